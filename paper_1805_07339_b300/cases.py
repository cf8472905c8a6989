"""Small, self-contained runs of single kernels, for profiling with ncu.

    python -m paper_1805_07339_b300.cases hist --frames 512 --reps 3
runs the fused hist+score kernel over the first `frames` frames of a 1080p
video generated on the device, `reps` times.  Sizes stay a few GB so that a
profiler capture ends by itself.
"""
from __future__ import annotations

import argparse


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("kernel", choices=["hist", "resize", "thumbs", "proposal", "cascade"])
    ap.add_argument("--frames", type=int, default=512)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--stride", type=int, default=1)
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--chunk-rows", type=int, default=0)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    a = ap.parse_args()
    import torch
    from . import scn
    from .workloads import MASTER_SEED
    W, H, T = a.width, a.height, a.frames
    fb = W * H * 3 // 2
    v = scn.scn_video_create(MASTER_SEED, 0, W, H, T, max(1, T // 120))
    buf = torch.empty(T * fb, dtype=torch.uint8, device="cuda")
    scn.scn_generate(v, buf, 0, T, fb)
    t = scn.scn_table_create(buf, W, H, T)
    seq = scn.scn_sample(t, scn.SCN_STRIDE, start=0, stop=T, step=a.stride)
    n = scn.scn_seq_length(seq)
    if a.grid or a.chunk_rows:
        scn.scn_seq_set_tune(seq, chunk_rows=a.chunk_rows, grid=a.grid)
    if a.kernel == "hist":
        h = torch.empty((n, 48), dtype=torch.int32, device="cuda")
        s = torch.empty(n, dtype=torch.int32, device="cuda")
        f = torch.empty(n, dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            scn.scn_hist_scores(seq, h, s, f)
    elif a.kernel == "resize":
        o = torch.empty((n, 3, 224, 224), dtype=torch.float32, device="cuda")
        for _ in range(a.reps):
            scn.scn_resize_norm(seq, 224, 224, (0.485, 0.456, 0.406), (0.229, 0.224, 0.225), scn.SCN_F32, o)
    elif a.kernel == "thumbs":
        o = torch.empty((n, 36, 64), dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            scn.scn_thumbs(seq, o)
    elif a.kernel == "cascade":
        # cascade proposal path with He-uniform weights: the difference prefilter at the
        # 98.5% quantile of this video's differences, the network threshold at its median
        from .proposal import he_uniform
        net = scn.scn_cnn_create(8)
        scn.scn_cnn_set_params(net, he_uniform(0))
        th = torch.empty((n, 36, 64), dtype=torch.uint8, device="cuda")
        d = torch.empty(n, dtype=torch.float32, device="cuda")
        z = torch.empty(max(n - 1, 1), dtype=torch.float32, device="cuda")
        scn.scn_thumbs(seq, th)
        scn.scn_thumb_diff(th, n, d)
        scn.scn_cnn_forward(net, th, n - 1, z)
        tau_d = float(torch.quantile(d[1:], 0.985).item())
        tau_n = float(torch.quantile(z[:n - 1], 0.5).item())
        g = torch.empty(n, dtype=torch.float32, device="cuda")
        pr = torch.empty(n, dtype=torch.uint8, device="cuda")
        sc = torch.empty(n, dtype=torch.int32, device="cuda")
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            scn.scn_cascade_hist_scores(seq, net, tau_d, tau_n, th, d, g, pr, sc, fl)
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        scn.scn_cnn_destroy(net)
    else:
        # learned proposal path with He-uniform weights and a threshold that
        # proposes about 1% of the pairs
        from .proposal import he_uniform
        net = scn.scn_cnn_create(4096)
        scn.scn_cnn_set_params(net, he_uniform(0))
        th = torch.empty((n, 36, 64), dtype=torch.uint8, device="cuda")
        z = torch.full((n,), -1e30, dtype=torch.float32, device="cuda")
        scn.scn_thumbs(seq, th)
        scn.scn_cnn_forward(net, th, n - 1, z[1:])
        tau = float(torch.quantile(z[1:], 0.99).item())
        pr = torch.empty(n, dtype=torch.uint8, device="cuda")
        sc = torch.empty(n, dtype=torch.int32, device="cuda")
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            scn.scn_proposal_hist_scores(seq, net, tau, th, z, pr, sc, fl)
        assert scn.scn_cnn_sync_status(net) == scn.SCN_OK
        scn.scn_cnn_destroy(net)
    torch.cuda.synchronize()
    assert scn.scn_seq_sync_status(seq) == scn.SCN_OK
    scn.scn_seq_destroy(seq)
    scn.scn_table_destroy(t)
    scn.scn_video_destroy(v)
    print(f"ok {a.kernel} frames={n}")


if __name__ == "__main__":
    main()
