"""Stream runner: many videos, only their sampled rows generated on the device in
bounded chunks, each chunk histogrammed and scored by one batched plan.

The paper streams a large video collection through its pipeline, decoding only
the frames a sampling op needs (Sec. 4.2, Sec. 4.3; STRIDED storage, Appendix
A.1); here the generator stands in for decode.  Every step runs in libscn's
kernels; this module groups videos into chunks, sequences the calls and keeps
the outputs.

Pipelining: all work goes on one CUDA stream; chunks alternate between two
device buffers, so the host prepares chunk c+1 (shot tables, tables, sequences,
plan) while the GPU still runs chunk c, and the stream order keeps chunk c+2's
generation behind chunk c's plan.  Library objects are released only at the
end (a device free would synchronise the device and stall the pipeline).
"""
from __future__ import annotations

import time

import numpy as np

from . import scn
from .workloads import MASTER_SEED


def sampled_rows(v: dict) -> np.ndarray:
    """Rows a video must materialise: the union of its stride and gather frames."""
    return np.union1d(v["stride"], v["gather"]).astype(np.int64)


def plan_chunks(spec: list[dict], chunk_bytes: int, rows_of: list | None = None) -> list[list[int]]:
    """Consecutive videos grouped so that each group's sampled rows fit chunk_bytes
    (rows_of: each video's sampled rows, when the caller has them already)."""
    chunks, cur, used = [], [], 0
    for i, v in enumerate(spec):
        nrows = len(rows_of[i]) if rows_of is not None else len(sampled_rows(v))
        need = nrows * (v["width"] * v["height"] * 3 // 2)
        if need > chunk_bytes:
            raise ValueError(f"video {v['video_id']} needs {need} bytes, more than a chunk")
        if cur and used + need > chunk_bytes:
            chunks.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += need
    if cur:
        chunks.append(cur)
    return chunks


class StreamResult:
    def __init__(self):
        self.videos = 0
        self.frames = 0          # sampled frames histogrammed (stride + gather sequences)
        self.nv12_bytes = 0      # NV12 bytes the plans read
        self.generated = 0       # rows generated
        self.chunks = 0
        self.ms_gen = 0.0        # device time of the generator launches
        self.ms_hist = 0.0       # device time of the plan launches
        self.ms_wall = 0.0
        self.stride = {}         # video index -> (score, flag) numpy arrays
        self.gather = {}
        self.hist = {}           # video index -> (stride hist, gather hist) for kept videos
        self.thumbs = {}         # video index -> stride-sequence thumbnails (when requested)

    def summary(self) -> dict:
        s = self.ms_wall / 1000
        return dict(videos=self.videos, frames=self.frames, chunks=self.chunks, nv12_GB=self.nv12_bytes / 1e9,
                    wall_s=s, frames_per_s=self.frames / s if s else 0.0,
                    hist_ms=self.ms_hist, hist_frames_per_s=self.frames / (self.ms_hist / 1000),
                    hist_GB_per_s=self.nv12_bytes / (self.ms_hist / 1000) / 1e9, gen_ms=self.ms_gen,
                    gen_GB_per_s=self.generated / (self.ms_gen / 1000) / 1e9 if self.ms_gen else 0.0)


def run_stream(torch, spec: list[dict], chunk_bytes: int = 4 << 30, tune: dict | None = None,
               keep_hist=(), thumbs: bool = False) -> StreamResult:
    """Generate, histogram and score every video of spec; returns scores and flags per
    video (and histograms for the video indices in keep_hist)."""
    if not spec:
        return StreamResult()
    W, H = spec[0]["width"], spec[0]["height"]
    if any(v["width"] != W or v["height"] != H for v in spec):
        raise ValueError("one frame size per stream")
    fb = W * H * 3 // 2
    # every video's row list, computed once and uploaded once (a per-video copy from
    # pageable memory could make the host wait for the stream)
    rows_of = [sampled_rows(v) for v in spec]
    chunks = plan_chunks(spec, chunk_bytes, rows_of)
    nbuf = 2 if len(chunks) > 1 else 1
    cap = max(sum(len(rows_of[i]) for i in c) for c in chunks) * fb
    bufs = [torch.empty(cap, dtype=torch.uint8, device="cuda") for _ in range(nbuf)]
    st = torch.cuda.Stream()
    keep_hist = set(keep_hist)
    row_off = np.concatenate([[0], np.cumsum([len(r) for r in rows_of])])
    d_rows_all = torch.from_numpy(np.concatenate(rows_of)).pin_memory().to("cuda")
    res = StreamResult()
    owned = dict(videos=[], tables=[], seqs=[], plans=[])
    outputs = []   # (chunk videos, per-video output tensors)
    events = []
    t0 = time.perf_counter()
    try:
        with torch.cuda.stream(st):
            for c, chunk in enumerate(chunks):
                buf = bufs[c % nbuf]
                off = 0
                seqs, hs, ss, fs, per_video = [], [], [], [], []
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                ev[0].record(st)
                for i in chunk:
                    v = spec[i]
                    rows = rows_of[i]
                    vid = scn.scn_video_create(MASTER_SEED, v["video_id"], W, H, v["num_frames"], 0, v["shot_mode"])
                    owned["videos"].append(vid)
                    d_rows = d_rows_all[row_off[i]:row_off[i + 1]]
                    scn.scn_generate_frames(vid, d_rows, buf[off:off + len(rows) * fb], fb, stream=st)
                    t = scn.scn_table_create(None, W, H, v["num_frames"], fb, rows=rows, d_nv12=buf.data_ptr() + off)
                    owned["tables"].append(t)
                    off += len(rows) * fb
                    s1 = scn.scn_sample(t, scn.SCN_STRIDE, 0, v["num_frames"], int(v["stride"][1] - v["stride"][0])
                                        if len(v["stride"]) > 1 else 1)
                    s2 = scn.scn_sample(t, scn.SCN_GATHER, indices=v["gather"])
                    owned["seqs"] += [s1, s2]
                    outs = []
                    for s_, n in ((s1, len(v["stride"])), (s2, len(v["gather"]))):
                        o = (torch.empty((n, 48), dtype=torch.int32, device="cuda"),
                             torch.empty(n, dtype=torch.int32, device="cuda"),
                             torch.empty(n, dtype=torch.uint8, device="cuda"))
                        seqs.append(s_)
                        hs.append(o[0])
                        ss.append(o[1])
                        fs.append(o[2])
                        outs.append(o)
                    th = None
                    if thumbs:
                        th = torch.empty((len(v["stride"]), 36, 64), dtype=torch.uint8, device="cuda")
                    per_video.append((i, outs, s1, th))
                    res.generated += len(rows) * fb
                    res.frames += len(v["stride"]) + len(v["gather"])
                ev[1].record(st)
                plan = scn.scn_plan_create(seqs, hs, ss, fs, tune)
                owned["plans"].append(plan)
                res.nv12_bytes += scn.scn_plan_info(plan)["nv12_bytes"]
                scn.scn_plan_run(plan, st)
                ev[2].record(st)
                if thumbs:
                    for _, _, s1, th in per_video:
                        scn.scn_thumbs(s1, th, st)
                events.append(ev)
                outputs.append(per_video)
                res.chunks += 1
        st.synchronize()
        res.ms_wall = (time.perf_counter() - t0) * 1000
        for p in owned["plans"]:
            if scn.scn_plan_sync_status(p, st) != scn.SCN_OK:
                raise RuntimeError("device status error in a stream plan")
        for ev in events:
            res.ms_gen += ev[0].elapsed_time(ev[1])
            res.ms_hist += ev[1].elapsed_time(ev[2])
        for per_video in outputs:
            for i, outs, _, th in per_video:
                (h1, s1_, f1), (h2, s2_, f2) = outs
                res.stride[i] = (s1_.cpu().numpy(), f1.cpu().numpy())
                res.gather[i] = (s2_.cpu().numpy(), f2.cpu().numpy())
                if i in keep_hist:
                    res.hist[i] = (h1.cpu().numpy(), h2.cpu().numpy())
                if th is not None:
                    res.thumbs[i] = th
        res.videos = len(spec)
        return res
    finally:
        for p in owned["plans"]:
            scn.scn_plan_destroy(p)
        for s_ in owned["seqs"]:
            scn.scn_seq_destroy(s_)
        for t in owned["tables"]:
            scn.scn_table_destroy(t)
        for v in owned["videos"]:
            scn.scn_video_destroy(v)
