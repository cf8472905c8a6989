"""The C ABI without a GPU: the library loads, exports every declared symbol,
and its host-only logic (argument checks, sampling, shot table) is right."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(scn_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1805_07339_b300 import scn
    lib = ctypes.CDLL(scn.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    bound = {n for n, _, _ in scn.SIGNATURES}
    assert declared == bound


def test_status_strings():
    from paper_1805_07339_b300 import scn
    for s in range(7):
        assert scn.lib().scn_status_str(s).decode()
    assert "unknown" in scn.lib().scn_status_str(99).decode()
    assert scn.scn_version().startswith("scn")


FAKE = 0x7F0000000000  # an aligned non-null address: tables never dereference on the host


def test_table_validation():
    from paper_1805_07339_b300 import scn
    t = scn.scn_table_create(None, 320, 180, 240, d_nv12=FAKE)
    scn.scn_table_destroy(t)
    bad = [dict(width=330, height=180), dict(width=320, height=181), dict(width=0, height=180)]
    for b in bad:
        with pytest.raises(scn.ScnError) as e:
            scn.scn_table_create(None, b["width"], b["height"], 10, d_nv12=FAKE)
        assert e.value.status == scn.SCN_EINVAL
    with pytest.raises(scn.ScnError):
        scn.scn_table_create(None, 320, 180, 10, d_nv12=FAKE + 8)  # misaligned
    with pytest.raises(scn.ScnError):
        scn.scn_table_create(None, 320, 180, 10, frame_stride=86400 + 8, d_nv12=FAKE)
    with pytest.raises(scn.ScnError):
        scn.scn_table_create(None, 320, 180, 10, rows=[3, 2], d_nv12=FAKE)
    with pytest.raises(scn.ScnError):
        scn.scn_table_create(None, 320, 180, 10, keyframes=[0, 10], d_nv12=FAKE)


def test_sampling_matches_oracle(orc):
    from paper_1805_07339_b300 import scn
    from tests.inputs import random_indices
    T = 7200
    kf = orc.Video(20180805, 0, 1920, 1080, T, num_shots=60).keyframes()
    t = scn.scn_table_create(None, 1920, 1080, T, keyframes=kf.tolist(), d_nv12=FAKE)
    try:
        cases = [
            (scn.SCN_STRIDE, dict(start=0, stop=T, step=1)),
            (scn.SCN_STRIDE, dict(start=0, stop=T, step=24)),
            (scn.SCN_STRIDE, dict(start=5, stop=100, step=7)),
            (scn.SCN_RANGE, dict(start=2000, stop=4000)),
            (scn.SCN_STRIDE, dict(start=10, stop=10, step=3)),
            (scn.SCN_GATHER, dict(indices=random_indices(1, T, 1000).tolist())),
            (scn.SCN_GATHER, dict(indices=[5, 5, 3, 7199, 0])),
            (scn.SCN_GATHER, dict(indices=[])),
            (scn.SCN_KEYFRAME, dict()),
        ]
        for kind, kw in cases:
            got = scn.scn_sample_indices(t, kind, **kw)
            ref = orc.sample(kind, T, keyframes=kf, **kw)
            assert got == ref.tolist(), (kind, kw)
        for kind, kw in [(scn.SCN_STRIDE, dict(start=0, stop=T + 1, step=1)),
                         (scn.SCN_STRIDE, dict(start=-1, stop=5, step=1)),
                         (scn.SCN_GATHER, dict(indices=[0, T]))]:
            with pytest.raises(scn.ScnError) as e:
                scn.scn_sample_indices(t, kind, **kw)
            assert e.value.status == scn.SCN_ERANGE
        with pytest.raises(scn.ScnError) as e:
            scn.scn_sample_indices(t, scn.SCN_STRIDE, start=0, stop=10, step=0)
        assert e.value.status == scn.SCN_EINVAL
    finally:
        scn.scn_table_destroy(t)


def test_sparse_table_rows():
    from paper_1805_07339_b300 import scn
    rows = list(range(0, 7200, 24))
    t = scn.scn_table_create(None, 640, 360, 7200, rows=rows, d_nv12=FAKE)
    try:
        assert scn.scn_sample_indices(t, scn.SCN_STRIDE, start=0, stop=7200, step=48) == list(range(0, 7200, 48))
        with pytest.raises(scn.ScnError) as e:
            scn.scn_sample_indices(t, scn.SCN_GATHER, indices=[24, 25])
        assert e.value.status == scn.SCN_ERANGE
    finally:
        scn.scn_table_destroy(t)


@pytest.mark.parametrize("W,H,T,S,mode", [(320, 180, 240, 8, 0), (1920, 1080, 7200, 60, 0),
                                          (640, 360, 54000, 0, 1), (64, 36, 3, 3, 0), (64, 36, 1, 1, 0)])
def test_shot_table_matches_oracle(orc, W, H, T, S, mode):
    from paper_1805_07339_b300 import scn
    for vid in (0, 1, 17):
        got = scn.scn_gen_shots(20180805, vid, W, H, T, num_shots=S, shot_mode=mode)
        ref = orc.Video(20180805, vid, W, H, T, num_shots=S, shot_mode=mode).shots()
        assert got == ref


def test_gen_params_rejected():
    from paper_1805_07339_b300 import scn
    for kw in [dict(width=330), dict(height=181), dict(num_frames=0), dict(num_shots=0), dict(num_shots=300)]:
        p = dict(width=320, height=180, num_frames=240, num_shots=8)
        p.update(kw)
        with pytest.raises(scn.ScnError):
            scn.scn_gen_shots(1, 0, p["width"], p["height"], p["num_frames"], p["num_shots"])


def test_autotune_cache_key_and_file(tmp_path, monkeypatch):
    from paper_1805_07339_b300 import autotune
    import numpy as np
    vids = [dict(width=640, height=360, sampling="stride1", frames=np.arange(100)),
            dict(width=1920, height=1080, sampling="gather5", frames=np.arange(7))]
    k1 = autotune.plan_key("B300", vids)
    k2 = autotune.plan_key("B300", list(reversed(vids)))
    assert k1 == k2 and "640x360:1" in k1 and "gather5:1" in k1
    calls = []
    monkeypatch.setattr(autotune.scn, "scn_plan_autotune",
                        lambda p, reps=3, stream=None: (calls.append(p) or ({"chunk_rows": 0, "grid": 0, "item_kpx": 2100}, 1.5)))
    applied = []
    monkeypatch.setattr(autotune.scn, "scn_plan_set_tune", lambda p, **t: applied.append(t))
    path = str(tmp_path / "c.json")
    r1 = autotune.tune_plan(7, k1, path)
    r2 = autotune.tune_plan(8, k1, path)
    assert not r1["cached"] and r2["cached"] and calls == [7] and applied == [r1["tune"]]
