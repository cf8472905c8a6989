"""Gated exact path and the learned proposal pipeline on the GPU: the exact
kernel has the final say on every proposed pair, unproposed pairs get 0."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from tests.inputs import MASTER_SEED, TINY  # noqa: E402


@pytest.fixture(scope="module")
def scn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07339_b300 import scn as s
    return s


@pytest.fixture(scope="module")
def tiny(scn):
    W, H, T, S = TINY["width"], TINY["height"], TINY["num_frames"], TINY["num_shots"]
    fb = W * H * 3 // 2
    v = scn.scn_video_create(MASTER_SEED, 0, W, H, T, S)
    buf = torch.empty(T * fb, dtype=torch.uint8, device="cuda")
    scn.scn_generate(v, buf, 0, T, fb)
    t = scn.scn_table_create(buf, W, H, T)
    seq = scn.scn_sample(t, scn.SCN_STRIDE, start=0, stop=T, step=1)
    h = torch.empty((T, 48), dtype=torch.int32, device="cuda")
    s = torch.empty(T, dtype=torch.int32, device="cuda")
    f = torch.empty(T, dtype=torch.uint8, device="cuda")
    scn.scn_hist_scores(seq, h, s, f)
    exact = (s.cpu().numpy().view(np.uint32).copy(), f.cpu().numpy().copy())
    yield dict(seq=seq, T=T, exact=exact, buf=buf)
    scn.scn_seq_destroy(seq)
    scn.scn_table_destroy(t)
    scn.scn_video_destroy(v)


def _outs(T):
    return (torch.empty(T, dtype=torch.uint8, device="cuda"), torch.full((T,), 7, dtype=torch.int32, device="cuda"),
            torch.full((T,), 7, dtype=torch.uint8, device="cuda"))


def _check(prop, sc, fl, exact):
    p = prop.cpu().numpy().astype(bool)
    s = sc.cpu().numpy().view(np.uint32)
    f = fl.cpu().numpy()
    es, ef = exact
    assert not p[0]
    assert np.array_equal(s[p], es[p]) and np.array_equal(f[p], ef[p])
    assert not s[~p].any() and not f[~p].any()
    return p


def test_gate_all_and_random(scn, tiny):
    T = tiny["T"]
    prop, sc, fl = _outs(T)
    gate = torch.ones(T, dtype=torch.float32, device="cuda")
    m = scn.scn_gated_hist_scores(tiny["seq"], gate, 0.0, prop, sc, fl)
    assert m == T - 1
    p = _check(prop, sc, fl, tiny["exact"])
    assert p[1:].all()
    rng = np.random.default_rng(1)
    g = rng.random(T).astype(np.float32)
    for tau in (0.5, 0.97, 2.0):
        m = scn.scn_gated_hist_scores(tiny["seq"], torch.from_numpy(g).cuda(), tau, prop, sc, fl)
        p = _check(prop, sc, fl, tiny["exact"])
        assert m == int(p.sum()) == int((g[1:] > tau).sum())


def test_gate_async_calls_in_a_row(scn, tiny):
    """Without the count the calls never wait for the GPU; back-to-back calls on one sequence (none,
    all, some proposed) each stay exact, so every device counter is left clean for the next."""
    T = tiny["T"]
    rng = np.random.default_rng(2)
    g_host = rng.random(T).astype(np.float32)
    g = torch.from_numpy(g_host).cuda()
    taus = (2.0, -1.0, 0.9, 0.3)
    outs = [_outs(T) for _ in taus]
    for (prop, sc, fl), tau in zip(outs, taus):
        assert scn.scn_gated_hist_scores(tiny["seq"], g, tau, prop, sc, fl, count=False) is None
    torch.cuda.synchronize()
    for (prop, sc, fl), tau in zip(outs, taus):
        p = _check(prop, sc, fl, tiny["exact"])
        assert int(p.sum()) == int((g_host[1:] > tau).sum())


def test_proposal_passes_in_a_row(scn, tiny):
    """Cascade, learned and gated passes queued back to back on one stream with no host wait
    (each pass's kernels are dependent launches; the list counters are zeroed inside the
    thumbnail and prefilter launches): every pass's outputs equal those of the same call made
    alone, with the device idle before and after it."""
    from paper_1805_07339_b300.proposal import he_uniform
    T = tiny["T"]
    net = scn.scn_cnn_create(64)
    try:
        scn.scn_cnn_set_params(net, he_uniform(5))
        th = torch.empty((T, 36, 64), dtype=torch.uint8, device="cuda")
        yuv = torch.empty((T, 3, 6, 32), dtype=torch.uint8, device="cuda")
        d = torch.empty(T, dtype=torch.float32, device="cuda")
        zz = torch.empty(T - 1, dtype=torch.float32, device="cuda")
        scn.scn_thumbs_yuv(tiny["seq"], th, yuv)
        scn.scn_thumb_diff_yuv(yuv, T, d)
        scn.scn_cnn_forward(net, th, T - 1, zz)
        dh, zh = d.cpu().numpy(), zz.cpu().numpy()
        g = torch.from_numpy(np.random.default_rng(9).random(T).astype(np.float32)).cuda()
        passes = [("cascade", float(np.quantile(dh[1:], 0.3)), float(np.quantile(zh, 0.4))),
                  ("learned", float(np.quantile(zh, 0.8)), None),
                  ("gated", 0.6, None),
                  ("cascade", float(np.quantile(dh[1:], 0.8)), float(np.quantile(zh, 0.1))),
                  ("learned", float(np.quantile(zh, 0.2)), None)]

        def run(kind, a, b, count):
            th_, yuv_, d_, gate = (torch.zeros_like(th), torch.zeros_like(yuv), torch.zeros_like(d),
                                   torch.full((T,), -1e30, dtype=torch.float32, device="cuda"))
            prop, sc, fl = _outs(T)
            if kind == "cascade":
                scn.scn_cascade_hist_scores(tiny["seq"], net, a, b, th_, yuv_, d_, gate, prop, sc, fl, count=count)
            elif kind == "learned":
                scn.scn_proposal_hist_scores(tiny["seq"], net, a, th_, gate, prop, sc, fl, count=count)
            else:
                scn.scn_gated_hist_scores(tiny["seq"], g, a, prop, sc, fl, count=count)
            return prop, sc, fl, gate

        alone = []
        for kind, a, b in passes:
            torch.cuda.synchronize()
            out = run(kind, a, b, True)
            torch.cuda.synchronize()
            _check(*out[:3], tiny["exact"])
            alone.append([x.cpu() for x in out])
        torch.cuda.synchronize()
        queued = [run(kind, a, b, False) for kind, a, b in passes]
        torch.cuda.synchronize()
        for (kind, _, _), q, ref in zip(passes, queued, alone):
            for x, y in zip(q, ref):
                assert torch.equal(x.cpu(), y), kind
        assert any(int(r[0].sum()) > 0 for r in alone)
        assert scn.scn_seq_sync_status(tiny["seq"]) == scn.SCN_OK
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
    finally:
        scn.scn_cnn_destroy(net)


def test_thumb_diff(scn, orc, tiny):
    T = tiny["T"]
    th = torch.empty((T, 36, 64), dtype=torch.uint8, device="cuda")
    scn.scn_thumbs(tiny["seq"], th)
    d = torch.empty(T, dtype=torch.float32, device="cuda")
    scn.scn_thumb_diff(th, T, d)
    t = th.cpu().numpy().astype(np.int64)
    ref = np.concatenate([[0.0], np.abs(np.diff(t, axis=0)).sum(axis=(1, 2)) / 2304.0])
    assert np.allclose(d.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)
    # a 4-byte-aligned (not 16-byte-aligned) array takes the narrow-load path: same values
    raw = torch.zeros(T * 2304 + 16, dtype=torch.uint8, device="cuda")
    off = raw[4:4 + T * 2304]
    off.copy_(th.reshape(-1))
    d4 = torch.empty(T, dtype=torch.float32, device="cuda")
    scn.scn_thumb_diff(off, T, d4)
    assert torch.equal(d4, d)


def test_thumb_diff_yuv_matches_oracle(scn, orc, tiny):
    """The luma + chroma difference gate over coarse YUV thumbnails against the oracle's, on the
    generated video and on random bytes (every sample difference up to 255)."""
    T = tiny["T"]
    yuv = torch.empty((T, 3, 6, 32), dtype=torch.uint8, device="cuda")
    scn.scn_thumbs_yuv(tiny["seq"], None, yuv)
    rng = np.random.default_rng(5)
    ryuv = rng.integers(0, 256, (8, 3, 6, 32), dtype=np.uint8)
    for y_np in (yuv.cpu().numpy(), ryuv):
        n = len(y_np)
        d = torch.empty(n, dtype=torch.float32, device="cuda")
        scn.scn_thumb_diff_yuv(torch.from_numpy(y_np).cuda(), n, d)
        ref = [0.0] + [orc.thumb_diff_yuv(y_np[k - 1], y_np[k]) for k in range(1, n)]
        assert np.allclose(d.cpu().numpy(), ref, rtol=1e-6, atol=1e-5)
    with pytest.raises(scn.ScnError):  # coarse thumbnails must be 16-byte aligned
        raw = torch.zeros(2 * 576 + 16, dtype=torch.uint8, device="cuda")
        scn.scn_thumb_diff_yuv(raw[4:4 + 2 * 576], 2, torch.empty(2, device="cuda"))


def test_learned_proposal_path_consistent(scn, tiny):
    from paper_1805_07339_b300.proposal import he_uniform
    T = tiny["T"]
    net = scn.scn_cnn_create(64)
    try:
        scn.scn_cnn_set_params(net, he_uniform(3))
        th = torch.empty((T, 36, 64), dtype=torch.uint8, device="cuda")
        z = torch.full((T,), -1e30, dtype=torch.float32, device="cuda")
        prop, sc, fl = _outs(T)
        zz = torch.empty(T - 1, dtype=torch.float32, device="cuda")
        scn.scn_thumbs(tiny["seq"], th)
        scn.scn_cnn_forward(net, th, T - 1, zz)
        tau = float(np.median(zz.cpu().numpy()))
        m = scn.scn_proposal_hist_scores(tiny["seq"], net, tau, th, z, prop, sc, fl)
        p = _check(prop, sc, fl, tiny["exact"])
        assert np.array_equal(z.cpu().numpy()[1:], zz.cpu().numpy())
        assert np.array_equal(p[1:], zz.cpu().numpy() > tau) and m == int(p.sum())
    finally:
        scn.scn_cnn_destroy(net)


@pytest.mark.parametrize("q_diff,q_net", [(0.5, 0.5), (0.0, 0.0), (1.1, 0.5), (0.2, 0.9), (0.9, 0.2)])
def test_cascade_matches_its_two_thresholds(scn, tiny, q_diff, q_net):
    """The cascade proposes exactly the pairs whose thumbnail difference and network
    logit both pass (thresholds at quantiles of the tiny video's own scores; 1.1 lists
    no pair at all); its gate holds the full forward's logits bit for bit on the listed
    pairs and -inf elsewhere; the exact kernel keeps the final say."""
    from paper_1805_07339_b300.proposal import he_uniform
    T = tiny["T"]
    net = scn.scn_cnn_create(64)
    try:
        scn.scn_cnn_set_params(net, he_uniform(3))
        th = torch.empty((T, 36, 64), dtype=torch.uint8, device="cuda")
        d = torch.empty(T, dtype=torch.float32, device="cuda")
        zz = torch.empty(T - 1, dtype=torch.float32, device="cuda")
        yuv = torch.empty((T, 3, 6, 32), dtype=torch.uint8, device="cuda")
        scn.scn_thumbs_yuv(tiny["seq"], th, yuv)
        scn.scn_thumb_diff_yuv(yuv, T, d)
        scn.scn_cnn_forward(net, th, T - 1, zz)
        dh, zh = d.cpu().numpy(), zz.cpu().numpy()
        tau_d = float(np.quantile(dh[1:], min(q_diff, 1.0))) + (1.0 if q_diff > 1.0 else 0.0)
        tau_n = float(np.quantile(zh, q_net))
        th2 = torch.zeros_like(th)
        d2 = torch.zeros_like(d)
        gate = torch.zeros(T, dtype=torch.float32, device="cuda")
        prop, sc, fl = _outs(T)
        yuv2 = torch.zeros_like(yuv)
        m = scn.scn_cascade_hist_scores(tiny["seq"], net, tau_d, tau_n, th2, yuv2, d2, gate, prop, sc, fl)
        p = _check(prop, sc, fl, tiny["exact"])
        assert torch.equal(yuv2, yuv)
        listed = np.concatenate([[False], dh[1:] > tau_d])
        want = listed & np.concatenate([[False], zh > tau_n])
        assert np.array_equal(p, want) and m == int(want.sum())
        assert np.array_equal(d2.cpu().numpy(), dh)
        # luma thumbnails written for both frames of every listed pair, nothing else
        frames = np.zeros(T, dtype=bool)
        frames[1:] |= dh[1:] > tau_d
        frames[:-1] |= dh[1:] > tau_d
        t2, t1 = th2.cpu().numpy(), th.cpu().numpy()
        assert np.array_equal(t2[frames], t1[frames]) and not t2[~frames].any()
        g = gate.cpu().numpy()
        assert np.array_equal(g[listed].view(np.uint32), np.concatenate([[0.0], zh]).astype(np.float32)[listed].view(np.uint32))
        assert np.all(np.isneginf(g[~listed]))
        assert scn.scn_seq_sync_status(tiny["seq"]) == scn.SCN_OK
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
    finally:
        scn.scn_cnn_destroy(net)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_cascade_short_sequences(scn, tiny, n):
    """0 elements: nothing written; 1: no pair, nothing proposed, no network launch;
    2-3: one or two pairs, each proposed exactly when both thresholds pass."""
    from paper_1805_07339_b300.proposal import he_uniform
    buf = tiny["buf"]
    W, H = 320, 180
    t = scn.scn_table_create(buf, W, H, tiny["T"])
    seq = scn.scn_sample(t, scn.SCN_STRIDE, start=10, stop=10 + n, step=1)
    net = scn.scn_cnn_create(8)
    try:
        scn.scn_cnn_set_params(net, he_uniform(4))
        m = max(n, 1)
        th = torch.full((m, 36, 64), 7, dtype=torch.uint8, device="cuda")
        yuv = torch.full((m, 3, 6, 32), 7, dtype=torch.uint8, device="cuda")
        d = torch.full((m,), 5.0, dtype=torch.float32, device="cuda")
        gate = torch.full((m,), 5.0, dtype=torch.float32, device="cuda")
        prop, sc, fl = (torch.full((m,), 9, dtype=torch.uint8, device="cuda"), torch.full((m,), 9, dtype=torch.int32, device="cuda"),
                        torch.full((m,), 9, dtype=torch.uint8, device="cuda"))
        cnt = scn.scn_cascade_hist_scores(seq, net, -1.0, -1e30, th, yuv, d, gate, prop, sc, fl)
        torch.cuda.synchronize()
        assert scn.scn_seq_sync_status(seq) == scn.SCN_OK
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        if n == 0:
            assert cnt == 0 and int(prop[0]) == 9 and float(gate[0]) == 5.0
            return
        # every difference passes -1 and every logit passes -1e30: all n-1 pairs proposed
        assert cnt == n - 1 and prop.cpu().numpy().tolist() == [0] + [1] * (n - 1)
        g = gate.cpu().numpy()
        assert np.isneginf(g[0]) and np.all(np.isfinite(g[1:]))
        h = torch.empty((n, 48), dtype=torch.int32, device="cuda")
        s2, f2 = torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda")
        scn.scn_hist_scores(seq, h, s2, f2)
        torch.cuda.synchronize()
        assert torch.equal(sc, s2) and torch.equal(fl, f2)
    finally:
        scn.scn_cnn_destroy(net)
        scn.scn_seq_destroy(seq)
        scn.scn_table_destroy(t)


def test_training_pipeline_small(scn):
    """A short GPU training run on two 1080p videos: the loss falls, the gated
    path stays exact on proposed pairs, and the report is complete."""
    from paper_1805_07339_b300 import proposal
    res = proposal.run(torch, steps=300, train_ids=[2000, 2001], val_ids=[3000], eval_ids=[4000])
    curve = res["train"]["curve"]
    assert curve[-1][1] < curve[0][1]
    for g in ("learned", "diff", "cascade"):
        assert res[g]["exact_on_proposed"]
        assert 0.0 <= res[g]["recall"] <= 1.0 and res[g]["speedup"] > 0
    assert res["boundaries"] > 0 and res["frames"] == 7200


def test_learned_gate_gains_over_thumbnail_difference(scn):
    """Full workload: train on 201,572 pairs (28 videos), pick thresholds on 8
    held-out videos, evaluate on 100,800 fresh 1080p frames.  The learned gate
    reaches >= 99% recall of the exact detector's boundaries and proposes fewer
    non-boundaries than the thumbnail-difference gate under the same rule; the
    cascade (luma + chroma difference prefilter, then the network) keeps >= 99.5%
    recall on this set and on two more sets of 14 fresh videos, and proposes far
    fewer pairs than the luma difference gate alone."""
    from paper_1805_07339_b300 import proposal
    res = proposal.run(torch, eval_sets=proposal.EVAL_SETS[1:])
    L, D = res["learned"], res["diff"]
    assert L["exact_on_proposed"] and D["exact_on_proposed"]
    assert L["recall"] >= 0.99
    assert L["precision"] > D["precision"]
    assert L["recall"] >= D["recall"]
    assert L["speedup"] > 1.0
    # the cascade (the difference gate as prefilter, the network as precision filter on what
    # it passes) keeps the target recall, proposes a subset of the difference gate's pairs,
    # and is more precise than it
    C = res["cascade"]
    assert C["exact_on_proposed"] and C["recall"] >= 0.995
    assert C["proposed"] <= D["proposed"] and C["precision"] > D["precision"]
    # the luma + chroma difference gate separates the held-out pairs with a margin, and the
    # cascade keeps its recall on each further set of 14 fresh videos
    V = res["val_cascade"]
    assert V["prefilter_recall"] == 1.0 and V["gate_lowest_boundary"] > V["gate_highest_non_boundary"]
    for e in res["eval_sets"]:
        assert e["cascade"]["recall"] >= 0.995 and e["boundaries"] > 700
    # and what the network gains: it removes most of the difference gate's proposals, i.e.
    # most of the exact re-reading (the end-to-end times of both gates are in the bench
    # record; a timing comparison does not belong in a correctness test)
    assert C["proposed"] < 0.75 * D["proposed"]
