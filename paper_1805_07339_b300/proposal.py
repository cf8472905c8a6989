"""The learned boundary proposal: data, training, threshold choice and evaluation.

Every number crunched here runs in libscn's kernels (generator, thumbnails,
exact histogram/score path, the network's forward/backward/Adam, the gated exact
path); this module only sequences the calls and counts.

Data (this library's reading of the proposal workload): 1080p synthetic videos of
7200 frames and 60 shots; a training pair is two consecutive frames (k-1, k)
labelled by the exact detector's flag of frame k.  Training, threshold and
evaluation videos use disjoint video ids.
"""
from __future__ import annotations

import time

import numpy as np

from . import scn
from .workloads import MASTER_SEED

HD = (1920, 1080, 7200, 60)
TRAIN_IDS = list(range(2000, 2028))     # 28 videos: 201,572 consecutive pairs
VAL_IDS = list(range(3000, 3008))       # threshold choice (~470 boundaries)
EVAL_IDS = list(range(4000, 4014))      # 14 x 7200 = 100,800 fresh frames
# two more disjoint evaluation sets of the same size: recall reported per set
EVAL_SETS = [EVAL_IDS, list(range(5000, 5014)), list(range(6000, 6014))]


def he_uniform(seed: int) -> np.ndarray:
    """Initial parameters: He-uniform weights (variance 2/fan_in), zero biases."""
    rng = np.random.default_rng(seed)
    shapes = [(16, 2, 3, 3), (16,), (32, 16, 3, 3), (32,), (32, 32, 3, 3), (32,), (64, 32), (64,), (1, 64), (1,)]
    out = []
    for sh in shapes:
        if len(sh) > 1:
            fan_in = int(np.prod(sh[1:]))
            out.append(rng.uniform(-1, 1, sh) * np.sqrt(6.0 / fan_in))
        else:
            out.append(np.zeros(sh))
    flat = np.concatenate([o.ravel() for o in out]).astype(np.float32)
    assert flat.size == scn.scn_cnn_num_params()
    return flat


class VideoSource:
    """Generates one synthetic 1080p video at a time into a reusable device buffer."""

    def __init__(self, torch, W=HD[0], H=HD[1], T=HD[2], S=HD[3]):
        self.torch, self.W, self.H, self.T, self.S = torch, W, H, T, S
        self.fb = W * H * 3 // 2
        self.buf = torch.empty(T * self.fb, dtype=torch.uint8, device="cuda")
        self.table = scn.scn_table_create(self.buf, W, H, T)
        self.seq = scn.scn_sample(self.table, scn.SCN_STRIDE, start=0, stop=T, step=1)
        t = torch
        self.hist = t.empty((T, 48), dtype=t.int32, device="cuda")
        self.score = t.empty(T, dtype=t.int32, device="cuda")
        self.flag = t.empty(T, dtype=t.uint8, device="cuda")

    def load(self, video_id: int) -> None:
        v = scn.scn_video_create(MASTER_SEED, video_id, self.W, self.H, self.T, self.S)
        scn.scn_generate(v, self.buf, 0, self.T, self.fb)
        scn.scn_video_destroy(v)

    def exact(self):
        scn.scn_hist_scores(self.seq, self.hist, self.score, self.flag)
        return self.flag

    def thumbs(self, out, yuv=None) -> None:
        scn.scn_thumbs_yuv(self.seq, out, yuv)

    def close(self) -> None:
        scn.scn_seq_destroy(self.seq)
        scn.scn_table_destroy(self.table)


def build_pairs(torch, src: VideoSource, ids: list[int], chroma: bool = False):
    """Thumbnails of every frame (and, with `chroma`, coarse YUV thumbnails), and
    (prev, cur, label) of every consecutive pair."""
    T = src.T
    thumbs = torch.empty((len(ids) * T, 36, 64), dtype=torch.uint8, device="cuda")
    uv = torch.empty((len(ids) * T, 3, 6, 32), dtype=torch.uint8, device="cuda") if chroma else None
    labels = []
    for i, vid in enumerate(ids):
        src.load(vid)
        src.thumbs(thumbs[i * T:(i + 1) * T], None if uv is None else uv[i * T:(i + 1) * T])
        labels.append(src.exact()[1:].float().clone())
    base = (torch.arange(len(ids), device="cuda") * T).repeat_interleave(T - 1)
    within = torch.arange(1, T, device="cuda").repeat(len(ids))
    cur = (base + within).int()
    prev = cur - 1
    if chroma:
        return thumbs, prev.contiguous(), cur.contiguous(), torch.cat(labels), uv
    return thumbs, prev.contiguous(), cur.contiguous(), torch.cat(labels)


def train(torch, net: int, thumbs, prev, cur, labels, steps: int = 2500, batch: int = 256, lr: float = 1e-3,
          seed: int = 0, log_every: int = 250, cosine: bool = True):
    """Adam on uniformly drawn batches of pairs; positive weight = negatives / positives;
    learning rate decayed to zero along a half cosine when `cosine` is set."""
    npos = float(labels.sum().item())
    pos_weight = (labels.numel() - npos) / max(npos, 1.0)
    rng = np.random.default_rng(seed)
    draws = torch.from_numpy(rng.integers(0, labels.numel(), (steps, batch)).astype(np.int64)).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    curve = []
    t0 = time.perf_counter()
    # every step's batch gathered up front, so that a step is the library's launches alone: one
    # chain of dependent launches, with no gather kernel and no loss copy except on logging steps
    bp_all = torch.index_select(prev, 0, draws.reshape(-1)).reshape(steps, batch)
    bc_all = torch.index_select(cur, 0, draws.reshape(-1)).reshape(steps, batch)
    by_all = torch.index_select(labels, 0, draws.reshape(-1)).reshape(steps, batch)
    for s in range(steps):
        lr_s = lr * 0.5 * (1.0 + np.cos(np.pi * s / steps)) if cosine else lr
        log = bool(log_every) and (s % log_every == 0 or s == steps - 1)
        scn.scn_cnn_train_step(net, thumbs, by_all[s], batch, pos_weight, max(lr_s, 1e-6), loss=loss if log else None,
                               prev=bp_all[s], cur=bc_all[s])
        if log:
            curve.append((s, float(loss.item())))
    torch.cuda.synchronize()
    return {"pos_weight": pos_weight, "steps": steps, "batch": batch, "lr": lr, "curve": curve,
            "seconds": time.perf_counter() - t0}


def logits(torch, net: int, thumbs, prev, cur):
    z = torch.empty(prev.numel(), dtype=torch.float32, device="cuda")
    scn.scn_cnn_forward(net, thumbs, prev.numel(), z, prev=prev, cur=cur)
    return z


def tau_for_recall(score: np.ndarray, labels: np.ndarray, recall: float = 0.99) -> float:
    """Largest threshold t with recall(score > t) >= recall on these labels."""
    pos = np.sort(score[labels > 0.5])
    if len(pos) == 0:
        return float("inf")
    keep = int(np.ceil(recall * len(pos)))  # positives that must score above t
    t = pos[len(pos) - keep]
    return float(np.nextafter(np.float32(t), np.float32(-np.inf)))


def choose_tau(score: np.ndarray, labels: np.ndarray, recall: float = 0.995, fp_rate: float = 1e-3) -> float:
    """Threshold picked on held-out pairs: low enough for `recall` of the
    positives, and further down to where the negatives' upper tail begins
    (their 1 - fp_rate quantile), since proposals below that cost almost nothing."""
    t_rec = tau_for_recall(score, labels, recall)
    neg = score[labels < 0.5]
    t_neg = float(np.quantile(neg, 1.0 - fp_rate)) if len(neg) else t_rec
    return min(t_rec, t_neg)


def evaluate(torch, net: int, tau: float, tau_diff: float, src: VideoSource, ids: list[int], reps: int = 3,
             tau_pre: float | None = None, tau_cascade: float | None = None, tau_yuv: float | None = None):
    """Per video: the plain exact path over all frames vs the learned gate, the
    luma thumbnail-difference gate, (when tau_yuv is given) the luma + chroma
    thumbnail-difference gate, and (when tau_pre is given) the cascade - the
    luma + chroma difference gate at tau_pre as prefilter, the network at
    tau_cascade on what passes - each as thumbnails + gate + exact path on
    proposed pairs."""
    T = src.T
    thumbs = torch.empty((T, 36, 64), dtype=torch.uint8, device="cuda")
    yuv = torch.empty((T, 3, 6, 32), dtype=torch.uint8, device="cuda")
    zl = torch.full((T,), -1e30, dtype=torch.float32, device="cuda")
    diff = torch.empty(T, dtype=torch.float32, device="cuda")
    prop = torch.empty(T, dtype=torch.uint8, device="cuda")
    sc = torch.empty(T, dtype=torch.int32, device="cuda")
    fl = torch.empty(T, dtype=torch.uint8, device="cuda")
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))  # noqa: E731
    tot = dict(frames=0, boundaries=0, t_plain=0.0)
    gates = ("learned", "diff") + (("diff_yuv",) if tau_yuv is not None else ()) + \
        (("cascade",) if tau_pre is not None else ())
    for gate in gates:
        tot[gate] = dict(tp=0, proposed=0, exact_equal=True)
        tot["t_" + gate] = 0.0
    for vid in ids:
        src.load(vid)
        torch.cuda.synchronize()
        exact = src.exact().clone()
        ex = exact.cpu().numpy()[1:].astype(bool)
        tot["frames"] += T
        tot["boundaries"] += int(ex.sum())
        # plain exact path
        a, b = ev()
        a.record()
        for _ in range(reps):
            src.exact()
        b.record()
        torch.cuda.synchronize()
        tot["t_plain"] += a.elapsed_time(b) / reps
        _check_status(src.seq, net, "plain exact path")
        for gate in gates:
            a, b = ev()
            a.record()
            for _ in range(reps):
                if gate == "learned":
                    scn.scn_proposal_hist_scores(src.seq, net, tau, thumbs, zl, prop, sc, fl, count=False)
                elif gate == "cascade":
                    scn.scn_cascade_hist_scores(src.seq, net, tau_pre, tau if tau_cascade is None else tau_cascade,
                                                thumbs, yuv, diff, zl, prop, sc, fl, count=False)
                elif gate == "diff_yuv":
                    src.thumbs(None, yuv)
                    scn.scn_thumb_diff_yuv(yuv, T, diff)
                    scn.scn_gated_hist_scores(src.seq, diff, tau_yuv, prop, sc, fl, count=False)
                else:
                    src.thumbs(thumbs)
                    scn.scn_thumb_diff(thumbs, T, diff)
                    scn.scn_gated_hist_scores(src.seq, diff, tau_diff, prop, sc, fl, count=False)
            b.record()
            torch.cuda.synchronize()
            tot["t_" + gate] += a.elapsed_time(b) / reps
            _check_status(src.seq, net, gate)
            p = prop.cpu().numpy()[1:].astype(bool)
            r = tot[gate]
            r["tp"] += int((p & ex).sum())
            r["proposed"] += int(p.sum())
            # the gated path reproduces the exact flag on every proposed pair
            fl_np = fl.cpu().numpy()[1:]
            r["exact_equal"] &= bool(np.array_equal(fl_np[p], ex[p].astype(np.uint8))) and not fl_np[~p].any()
    out = {"frames": tot["frames"], "boundaries": tot["boundaries"], "t_plain_ms": tot["t_plain"]}
    for gate in gates:
        r = tot[gate]
        out[gate] = {"recall": r["tp"] / max(tot["boundaries"], 1), "precision": r["tp"] / max(r["proposed"], 1),
                     "proposed": r["proposed"], "t_ms": tot["t_" + gate],
                     "speedup": tot["t_plain"] / max(tot["t_" + gate], 1e-9), "exact_on_proposed": r["exact_equal"]}
    return out


def _check_status(seq, net, where: str) -> None:
    """A bounded device wait that ran out would otherwise show only as stale
    scores: read both status words after every timed loop."""
    if scn.scn_seq_sync_status(seq) != scn.SCN_OK:
        raise RuntimeError(f"device timeout in the hist kernel ({where})")
    if scn.scn_cnn_sync_status(net) != scn.SCN_OK:
        raise RuntimeError(f"device timeout in the proposal network ({where})")


def run(torch, steps: int = 6000, batch: int = 256, lr: float = 1e-3, seed: int = 0, train_ids=None, val_ids=None,
        eval_ids=None, eval_sets=None) -> dict:
    """Build data, train on the GPU, pick thresholds on held-out videos (choose_tau),
    evaluate on eval_ids (the headline figures), and the cascade's recall and
    precision on each further set of eval_sets."""
    src = VideoSource(torch)
    try:
        th, pv, cu, lab = build_pairs(torch, src, train_ids or TRAIN_IDS)
        net = scn.scn_cnn_create(batch)
        fwd = scn.scn_cnn_create(4096)
        try:
            scn.scn_cnn_set_params(net, he_uniform(seed))
            tr = train(torch, net, th, pv, cu, lab, steps=steps, batch=batch, lr=lr, seed=seed)
            scn.scn_cnn_set_params(fwd, scn.scn_cnn_get_params(net))
            del th, pv, cu
            vth, vp, vc, vl, vuv = build_pairs(torch, src, val_ids or VAL_IDS, chroma=True)
            z = logits(torch, fwd, vth, vp, vc).cpu().numpy()
            vlab = vl.cpu().numpy()
            tau = choose_tau(z, vlab)
            d = torch.empty(vth.shape[0], dtype=torch.float32, device="cuda")
            # gate of pair (k-1, k) sits at thumbnail k; pairs never span two videos
            scn.scn_thumb_diff(vth, vth.shape[0], d)
            dv = d.cpu().numpy()[vc.cpu().numpy()]
            tau_d = choose_tau(dv, vlab)
            scn.scn_thumb_diff_yuv(vuv, vth.shape[0], d)
            dyv = d.cpu().numpy()[vc.cpu().numpy()]
            tau_yuv = choose_tau(dyv, vlab)
            # cascade: the luma + chroma difference gate as the prefilter (a boundary moves luma or
            # chroma, so boundaries and non-boundaries separate there, where the luma gate's
            # non-boundaries crowd just below the boundaries of chroma-dominant cuts), then the
            # network as a precision filter on what passes, with a threshold 2 logits below the
            # lowest held-out boundary there (and never stricter than the network's own)
            tau_pre = tau_yuv
            pas = dyv > tau_pre
            tau_c = min(tau_for_recall(z[pas], vlab[pas], recall=1.0) - 2.0, tau) if pas.any() else tau
            pos = vlab > 0.5
            neg = ~pos
            val_cascade = {"recall": float(np.mean(pas[pos] & (z[pos] > tau_c))), "prefilter_pass": float(np.mean(pas)),
                           "proposed_fraction": float(np.mean(pas & (z > tau_c))),
                           "prefilter_recall": float(np.mean(pas[pos])),
                           # the margin between the classes on the held-out gate values
                           "gate_lowest_boundary": float(dyv[pos].min()) if pos.any() else None,
                           "gate_highest_non_boundary": float(dyv[neg].max()) if neg.any() else None}
            res = evaluate(torch, fwd, tau, tau_d, src, eval_ids or EVAL_IDS, tau_pre=tau_pre, tau_cascade=tau_c,
                           tau_yuv=tau_yuv)
            sets = []
            for ids in (eval_sets or []):
                r2 = evaluate(torch, fwd, tau, tau_d, src, ids, reps=1, tau_pre=tau_pre, tau_cascade=tau_c,
                              tau_yuv=tau_yuv)
                sets.append({"videos": [ids[0], ids[-1]], "boundaries": r2["boundaries"],
                             **{g: {k: r2[g][k] for k in ("recall", "precision", "speedup")}
                                for g in ("cascade", "learned", "diff", "diff_yuv")}})
            res.update({"train": tr, "tau": tau, "tau_diff": tau_d, "tau_pre": tau_pre, "tau_cascade": tau_c,
                        "tau_yuv": tau_yuv, "val_cascade": val_cascade, "eval_sets": sets,
                        "train_pairs": int(lab.numel()),
                        "train_positives": int(lab.sum().item()), "val_pairs": int(vl.numel()),
                        "params": scn.scn_cnn_get_params(fwd)})
            return res
        finally:
            scn.scn_cnn_destroy(net)
            scn.scn_cnn_destroy(fwd)
    finally:
        src.close()


# ---------------------------------------------------------------------------
# The news-archive stream: a second model for stride-24 pairs of 640x360 videos
# ---------------------------------------------------------------------------
# Pairs 24 frames apart see a drifted ramp and, with geometric shots of mean
# length ~65, cross a boundary about a third of the time: a different input
# distribution from consecutive 1080p frames, so the stream gets its own model,
# trained and thresholded on stream-shaped videos with ids disjoint from the stream.
STREAM_TRAIN = dict(nvideos=160, seed=21, id0=400000)
STREAM_VAL = dict(nvideos=40, seed=22, id0=410000)


def stream_pairs(torch, spec: list[dict], res):
    """Concatenated thumbnails of every video's stride sequence and the (prev, cur,
    label) of its consecutive stride pairs (label = exact flag of the later frame)."""
    ths, prev, cur, lab = [], [], [], []
    off = 0
    for i in range(len(spec)):
        th = res.thumbs[i]
        n = th.shape[0]
        ths.append(th)
        k = torch.arange(1, n, device="cuda", dtype=torch.int32) + off
        prev.append(k - 1)
        cur.append(k)
        lab.append(torch.from_numpy(res.stride[i][1][1:].astype(np.float32)))
        off += n
    return torch.cat(ths), torch.cat(prev), torch.cat(cur), torch.cat(lab).cuda()


def run_stream_proposal(torch, eval_spec=None, steps: int = 3000, batch: int = 256, lr: float = 1e-3,
                        seed: int = 0) -> dict:
    """Train on stride-24 pairs of stream-shaped videos, pick tau on held-out ones, then
    score every stride-24 pair of the stream and compare with the exact flags."""
    from . import stream
    from .workloads import stream_spec
    tr_spec, va_spec = stream_spec(**STREAM_TRAIN), stream_spec(**STREAM_VAL)
    ev_spec = eval_spec if eval_spec is not None else stream_spec()
    net = scn.scn_cnn_create(batch)
    fwd = scn.scn_cnn_create(8)
    try:
        tr = stream.run_stream(torch, tr_spec, thumbs=True)
        th, pv, cu, lab = stream_pairs(torch, tr_spec, tr)
        del tr
        scn.scn_cnn_set_params(net, he_uniform(seed))
        trn = train(torch, net, th, pv, cu, lab, steps=steps, batch=batch, lr=lr, seed=seed, log_every=0)
        scn.scn_cnn_set_params(fwd, scn.scn_cnn_get_params(net))
        n_train, pos_train = int(lab.numel()), int(lab.sum().item())
        del th, pv, cu, lab
        va = stream.run_stream(torch, va_spec, thumbs=True)
        vth, vp, vc, vl = stream_pairs(torch, va_spec, va)
        del va
        tau = choose_tau(logits(torch, fwd, vth, vp, vc).cpu().numpy(), vl.cpu().numpy())
        del vth, vp, vc, vl
        ev = stream.run_stream(torch, ev_spec, thumbs=True)
        eth, ep, ec, el = stream_pairs(torch, ev_spec, ev)
        del ev
        z = torch.empty(ep.numel(), dtype=torch.float32, device="cuda")
        scn.scn_cnn_forward(fwd, eth, ep.numel(), z, prev=ep, cur=ec)  # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        scn.scn_cnn_forward(fwd, eth, ep.numel(), z, prev=ep, cur=ec)
        e1.record()
        torch.cuda.synchronize()
        if scn.scn_cnn_sync_status(fwd) != scn.SCN_OK:
            raise RuntimeError("device status error in the proposal network")
        p = (z.cpu().numpy() > tau)
        y = el.cpu().numpy() > 0.5
        tp = int((p & y).sum())
        return {"pairs": int(y.size), "positives": int(y.sum()), "proposed": int(p.sum()),
                "recall": tp / max(int(y.sum()), 1), "precision": tp / max(int(p.sum()), 1),
                "proposed_fraction": float(p.mean()), "tau": tau, "forward_ms": e0.elapsed_time(e1),
                "forward_pairs_per_s": y.size / (e0.elapsed_time(e1) / 1000),
                "train_pairs": n_train, "train_positives": pos_train, "train_steps": trn["steps"],
                "train_seconds": trn["seconds"]}
    finally:
        scn.scn_cnn_destroy(net)
        scn.scn_cnn_destroy(fwd)
